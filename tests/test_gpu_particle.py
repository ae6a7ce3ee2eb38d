"""GPU parity of the coupled step (collide+stream, 6DOF, stress, force and
torque, IBM cycles, window slide) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_15115_gb300 import inputs as I

from cases import TOL_U_F32, gpu_velocity, make_pair, rel_max

pytestmark = pytest.mark.gpu


def _compare_state(t, s, tol_f=1e-4, tol_v=1e-5, r0=None):
    a, b = t.state(), s.state()
    scale_f = max(np.abs(b["F"]).max(), 1e-300)
    assert np.abs(a["F"] - b["F"]).max() / scale_f < tol_f, (a["F"], b["F"])
    # the pressure part of the force (isotropic part of Eq. 10) alike
    assert np.abs(a["Fp"] - b["Fp"]).max() / max(scale_f, np.abs(b["Fp"]).max()) < tol_f, (a["Fp"], b["Fp"])
    scale_v = max(np.abs(b["v"]).max(), 1e-300)
    assert np.abs(a["v"] - b["v"]).max() / scale_v < tol_v, (a["v"], b["v"])
    # the position integrates v: the velocity tolerance times the distance travelled
    travelled = float(np.abs(b["r"] - r0).max()) if r0 is not None else 0.0
    assert np.abs(a["r"] - b["r"]).max() < 1e-6 + tol_v * travelled
    assert np.array_equal(a["origin"], b["origin"].astype(np.int64))
    return a, b


def test_sphere_in_closed_box_100_steps():
    # 32x32x64 closed box, sphere d = 8 (252 markers), kappa 2.5, g along -z,
    # seeded smooth random initial flow of amplitude 0.01
    shape = (64, 32, 32)
    V, T = I.sphere(5, 8.0)
    fields = I.random_state(shape, u_amp=0.01, rho_amp=0.001, kmax=4, seed=1)
    t, s = make_pair(32, 32, 64, 0.05, (1, 1, 1, 1), kappa=2.5, g=(0, 0, -1e-5), fields=fields,
                     particle=(V, T, (15.5, 15.5, 44.0), (0, 0, 0), (0, 0, 0)))
    _compare_state(t, s)
    t.step(100)
    s.step(100)
    u, _ = gpu_velocity(t)
    err = rel_max(u, s.velocity())
    assert err < TOL_U_F32, err
    _compare_state(t, s)


def test_tilted_ellipsoid_rotation_and_torque():
    shape = (48, 40, 40)
    V, T = I.ellipsoid(6, (6.0, 3.0, 3.0))
    V = I.rotate(I.rotate(V, "x", 30.0), "z", 20.0)
    fields = I.random_state(shape, u_amp=0.02, rho_amp=0.001, kmax=3, seed=2)
    t, s = make_pair(40, 40, 48, 0.04, (0, 0, 1, 2), kappa=2.0, g=(0, 0, -1e-4), sponge=6, fields=fields,
                     particle=(V, T, (19.7, 20.2, 22.3), (0, 0, -0.01), (0.002, -0.001, 0.003)))
    t.step(100)
    s.step(100)
    a, b = _compare_state(t, s, tol_f=1e-4, tol_v=1e-5)
    assert np.abs(a["w"] - b["w"]).max() / np.abs(b["w"]).max() < 1e-4
    assert np.abs(a["T"] - b["T"]).max() / np.abs(b["T"]).max() < 1e-3
    assert np.abs(a["d"] - b["d"]).max() < 1e-6
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < TOL_U_F32


def test_sliding_window_follows_particle():
    # falling sphere in a periodic column with the ring window; several slides
    shape = (48, 24, 24)
    V, T = I.sphere(4, 6.0)
    t, s = make_pair(24, 24, 48, 0.05, (0, 0, 1, 2), kappa=2.0, g=(0, 0, -2e-4), sponge=6, slide=1, anchor=0.5,
                     particle=(V, T, (11.6, 12.3, 24.4), (0, 0, -0.08), (0, 0, 0)))
    t.step(80)
    s.step(80)
    a, b = _compare_state(t, s, tol_f=1e-4, tol_v=1e-5, r0=np.array([11.6, 12.3, 24.4]))
    assert b["origin"][2] <= -2  # the window moved (the first slide wraps the ring index)
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < TOL_U_F32


def test_determinism_and_graph_equivalence():
    # two runs with the pipelined 8-step graphs (30 = 3 x 8 + 6 one-step
    # graphs), one with direct launches, one stepping one graph at a time
    V, T = I.sphere(4, 6.0)
    runs = []
    for flags, one in (({}, False), ({}, False), ({"no_graph": 1}, False), ({}, True)):
        t, _ = make_pair(24, 24, 32, 0.05, (0, 0, 1, 2), kappa=2.0, g=(0, 0, -1e-4), sponge=4, flags=flags,
                         particle=(V, T, (11.6, 12.3, 16.4), (0, 0, 0), (0, 0.001, 0)))
        if one:
            for _ in range(30):
                t.step(1)
        else:
            t.step(30)
        runs.append((t.populations().cpu().numpy(), t.state()))
    for other in runs[1:]:
        assert np.array_equal(runs[0][0], other[0])
        assert np.array_equal(runs[0][1]["F"], other[1]["F"])


def test_domain_error_is_latched_not_faulted():
    # a particle driven into the closed bottom face: the device latches EDOMAIN
    V, T = I.sphere(3, 4.0)
    t, _ = make_pair(16, 16, 16, 0.05, (1, 1, 1, 1), kappa=2.0, g=(0, 0, 0),
                     particle=(V, T, (8.0, 8.0, 5.2), (0, 0, -0.3), (0, 0, 0)))
    t.step(12)
    st = t.state(check=False)
    assert st["rc"] == 7 and st["status"] == 7


@pytest.mark.slow
def test_stokes_settling_cfg1_drag_and_velocity_vs_oracle():
    # the 32x32x64 sphere case for 500 steps: drag and settling velocity <= 0.5%
    V, T = I.sphere(5, 8.0)
    O.set_threads(0)
    t, s = make_pair(32, 32, 64, 0.05, (1, 1, 1, 1), kappa=2.5, g=(0, 0, -1e-5),
                     particle=(V, T, (15.5, 15.5, 44.0), (0, 0, 0), (0, 0, 0)))
    t.step(500)
    s.step(500)
    a, b = t.state(), s.state()
    assert abs(a["F"][2] - b["F"][2]) / abs(b["F"][2]) < 5e-3
    assert abs(a["v"][2] - b["v"][2]) / abs(b["v"][2]) < 5e-3


def test_held_sphere_in_shear_flow_vs_oracle():
    # a sphere with its centre held in the shear between two moving walls:
    # force, torque and the spin-up of its rotation against the oracle
    n = 24
    V, T = I.sphere(4, 6.0)
    z = np.arange(n) + 0.5
    u = np.zeros((n, n, n, 3))
    u[..., 0] = (-0.01 + 0.02 * z / n)[:, None, None]
    t, s = make_pair(n, n, n, 0.1, (0, 0, 3, 3), kappa=2.0, g=(0, 0, -1e-5), flags={"fixed_position": 1},
                     fields=(None, u), walls=((-0.01, 0, 0), (0.01, 0, 0)),
                     particle=(V, T, (11.6, 11.3, 11.8), (0, 0, 0), (0, 0, 0)))
    t.step(60)
    s.step(60)
    a, b = _compare_state(t, s)
    assert np.array_equal(a["v"], np.zeros(3)) and np.abs(a["r"] - np.array([11.6, 11.3, 11.8])).max() < 1e-12
    assert np.abs(a["w"] - b["w"]).max() < 1e-4 * np.abs(b["w"]).max()
    assert np.abs(a["T"] - b["T"]).max() < 1e-4 * np.abs(b["T"]).max()


def test_sphere_spin_up_in_shear_flow_follows_feuillebois_lasek():
    # the free-rotation validation: a sphere (d = 8, 252 markers) held at the
    # centre of a 48^3 box whose bottom and top walls move at -U and +U in x
    # (shear rate G = 2U/H, Re_G = 4 G r^2 / nu ~ 0.26), released from rest in
    # the fully developed shear: its angular velocity about y rises to the
    # fluid's G/2 along the unsteady-Stokes response of Eq. B.2 (a sudden
    # torque on a sphere at rest, normalised by its terminal value)
    from paper_2408_15115_gb300 import analysis as A
    from paper_2408_15115_gb300 import turret as Tu
    n, U, nu, kappa = 48, 0.01, 0.1, 2.0
    V, T = I.sphere(5, 8.0)
    t = Tu.Turret(n, n, n, nu, kappa, (0, 0, 0), 0, 0, 3, 3, flags={"fixed_position": 1})
    t.set_wall_velocity((-U, 0, 0), (U, 0, 0))
    z = np.arange(n) + 0.5
    u = np.zeros((n, n, n, 3))
    u[..., 0] = (-U + 2 * U * z / n)[:, None, None]
    t.set_fields(None, u)
    t.load_surface(V, T, (n / 2 - 0.5, n / 2 - 0.5, n / 2 - 0.5))
    wf = U / n  # G / 2
    ts, w = [], []
    for k in range(150):
        t.step(20)
        st = t.state()
        ts.append(20 * (k + 1))
        w.append(st["w"])
    w = np.array(w) / wf
    r = (3.0 * st["volume"] / (4.0 * np.pi)) ** (1.0 / 3.0)
    model = A.fl78_rotation_exact(r, nu, kappa, 1.0, np.array(ts)) * 8.0 * np.pi * nu * r ** 3
    t.close()
    print("w_y / (G/2) at t = 20, 100, 3000: %.4f %.4f %.4f; model %.4f %.4f %.4f" %
          (w[0, 1], w[4, 1], w[-1, 1], model[0], model[4], model[-1]))
    assert abs(w[-1, 1] - 1.0) < 1e-2            # terminal: the fluid's rotation rate G/2
    assert np.abs(w[:, 1] - model).max() < 0.05  # the spin-up follows Eq. B.2
    assert np.abs(w[:, [0, 2]]).max() < 1e-3     # about y only


@pytest.mark.parametrize("storage,tol_f,tol_v", [("f32", 1e-4, 1e-5), ("f16", 2e-2, 2e-3)])
def test_reinjection_copy_vs_oracle(storage, tol_f, tol_v):
    # the re-injection copy of Sec. 2.5: a falling sphere crosses the trigger
    # plane and the block of fluid around it is copied up with it; the window
    # origin, the trajectory and the force against the oracle through the event
    V, T = I.icosphere(3, 3.0)
    t, s = make_pair(16, 16, 64, 0.1, (0, 0, 1, 2), kappa=2.0, g=(0, 0, -1e-4), sponge=4, storage=storage,
                     reinject=(22, 40, 12, 14), particle=(V, T, (7.8, 8.1, 22.5), (0, 0, -0.05), (0, 0, 0)))
    t.step(60)
    s.step(60)
    a, b = _compare_state(t, s, tol_f=tol_f, tol_v=tol_v, r0=np.array([7.8, 8.1, 22.5]))
    assert a["origin"][2] < 0  # re-injected once: the window moved down
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < (TOL_U_F32 if storage == "f32" else 2e-3)

