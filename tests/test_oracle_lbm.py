"""Pins of the oracle's lattice, equilibrium, regularized collision and streaming.

Each pin checks the oracle against something other than itself: exact lattice
moments, the tensor-product closed form of the D3Q27 equilibrium, moment
identities of Appendix A, a brute-force pair sum for the a_1 recursion, the
decay rate of a Taylor-Green mode and the Poiseuille profile.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O

RNG = np.random.default_rng(1234)


def test_lattice_moments_exact():
    # Sec. 2.1 lattice with standard tensor-product weights (reading: weights not printed)
    xi, w = O.lattice()
    assert sorted(map(tuple, xi)) == sorted(itertools.product((-1, 0, 1), repeat=3))
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * xi).sum(0)).max() < 1e-16
    M2 = np.einsum("i,ia,ib->ab", w, xi, xi)
    assert np.abs(M2 - np.eye(3) / 3.0).max() < 1e-15
    assert abs((w * xi[:, 0] ** 4).sum() - 1.0 / 3.0) < 1e-15
    assert abs((w * xi[:, 0] ** 2 * xi[:, 1] ** 2).sum() - 1.0 / 9.0) < 1e-15
    assert abs((w * xi[:, 0] ** 2 * xi[:, 1] ** 2 * xi[:, 2] ** 2).sum() - 1.0 / 27.0) < 1e-15
    # opposite direction is 26 - i
    assert np.all(xi[::-1] == -xi)


def test_hermite_tensors_textbook():
    # H2_ab = xi_a xi_b - cs2 d_ab, H3_xxy = (xi_x^2 - cs2) xi_y, H4_xxyy = (xi_x^2-cs2)(xi_y^2-cs2)
    xi, w = O.lattice()
    cs2 = 1.0 / 3.0
    for i in range(27):
        x, y, z = xi[i]
        assert abs(O.hermite(i, [0, 0]) - (x * x - cs2)) < 1e-15
        assert abs(O.hermite(i, [0, 1]) - x * y) < 1e-15
        assert abs(O.hermite(i, [0, 0, 1]) - (x * x - cs2) * y) < 1e-15
        assert abs(O.hermite(i, [0, 1, 2]) - x * y * z) < 1e-15
        assert abs(O.hermite(i, [0, 0, 1, 1]) - (x * x - cs2) * (y * y - cs2)) < 1e-15
        assert abs(O.hermite(i, [0, 0, 1, 1, 2, 2]) - (x * x - cs2) * (y * y - cs2) * (z * z - cs2)) < 1e-15
        # 1-D Hermite He4 on a single axis: xi^4 - 6 cs2 xi^2 + 3 cs2^2
        assert abs(O.hermite(i, [0, 0, 0, 0]) - (x ** 4 - 6 * cs2 * x * x + 3 * cs2 * cs2)) < 1e-15


def _feq_product(rho, u):
    # closed form: rho prod_a w1(xi_a) [1 + 3 xi_a u_a + 9/2 (xi_a^2 - 1/3) u_a^2]
    xi, _ = O.lattice()
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
    out = np.zeros(27)
    for i in range(27):
        p = rho
        for a in range(3):
            e = xi[i][a]
            p *= w1[e] * (1 + 3 * e * u[a] + 4.5 * (e * e - 1.0 / 3.0) * u[a] ** 2)
        out[i] = p
    return out


@pytest.mark.parametrize("trial", range(6))
def test_feq_equals_product_form_and_moments(trial):
    rho = 1.0 + 0.05 * RNG.standard_normal()
    u = 0.1 * RNG.standard_normal(3)
    f0 = O.feq(rho, u)
    assert np.abs(f0 - _feq_product(rho, u)).max() < 2e-16 * 8
    xi, _ = O.lattice()
    assert abs(f0.sum() - rho) < 1e-14
    assert np.abs((f0[:, None] * xi).sum(0) - rho * u).max() < 1e-15
    M2 = np.einsum("i,ia,ib->ab", f0, xi, xi)
    assert np.abs(M2 - rho * (np.eye(3) / 3 + np.outer(u, u))).max() < 1e-15


def _a1_pairs(idx, P, u):
    # closed form of the recursion: sum over index pairs of P_{ij} times the other velocities
    tot = 0.0
    n = len(idx)
    for i in range(n):
        for j in range(i + 1, n):
            p = P[idx[i], idx[j]]
            for k in range(n):
                if k not in (i, j):
                    p *= u[idx[k]]
            tot += p
    return tot


def test_a1_recursion_matches_pair_sum():
    for _ in range(20):
        A = RNG.standard_normal((3, 3))
        P = A + A.T
        u = RNG.standard_normal(3)
        for n in (2, 3, 4, 5, 6):
            for idx in itertools.product(range(3), repeat=n):
                ref = _a1_pairs(idx, P, u)
                assert abs(O.a1(idx, P, u) - ref) < 1e-12 * max(1.0, abs(ref))


def test_fone_moments_and_idempotence():
    xi, _ = O.lattice()
    for _ in range(5):
        A = 1e-3 * RNG.standard_normal((3, 3))
        P = A + A.T
        u = 0.05 * RNG.standard_normal(3)
        f1 = O.fone(P, u)
        assert abs(f1.sum()) < 1e-17
        assert np.abs((f1[:, None] * xi).sum(0)).max() < 1e-17
        assert np.abs(np.einsum("i,ia,ib->ab", f1, xi, xi) - P).max() < 1e-17
        # regularization is a projection: moments of f0 + f1 give back P and f1
        rho = 1.01
        f = O.feq(rho, u) + f1
        r2, u2, P2 = O.moments(f)
        assert abs(r2 - rho) < 1e-15 and np.abs(u2 - u).max() < 1e-15
        # P2 carries the rounding of rho/3 (an O(1) quantity): a few ulp of 1
        assert np.abs(P2 - P).max() < 1e-15
        assert np.abs(O.fone(P2, u2) - f1).max() < 1e-15


def _random_f():
    rho = 1.0 + 0.01 * RNG.standard_normal()
    u = 0.03 * RNG.standard_normal(3)
    return O.feq(rho, u) + 1e-3 * O.lattice()[1] * RNG.standard_normal(27)


@pytest.mark.parametrize("scheme", [0, 1])
def test_collision_invariants(scheme):
    xi, _ = O.lattice()
    for tau in (0.51, 0.65, 1.0, 1.7):
        f = _random_f()
        rho, u, P = O.moments(f)
        out = O.collide_cell(f, np.zeros(3), tau, scheme)
        assert abs(out.sum() - f.sum()) < 1e-15
        assert np.abs((out[:, None] * xi).sum(0) - (f[:, None] * xi).sum(0)).max() < 1e-16
        M2 = np.einsum("i,ia,ib->ab", out, xi, xi)
        expect = rho * (np.eye(3) / 3 + np.outer(u, u)) + (1 - 1 / tau) * P
        assert np.abs(M2 - expect).max() < 1e-15
        h = 1e-4 * RNG.standard_normal(3)
        out = O.collide_cell(f, h, tau, scheme)
        gain = (out[:, None] * xi).sum(0) - (f[:, None] * xi).sum(0)
        want = rho * h if scheme == 0 else tau * rho * h
        assert np.abs(gain - want).max() < 1e-16
        assert abs(out.sum() - f.sum()) < 1e-15


def test_stress_formula():
    # Eq. 10 for an f whose off-equilibrium part is known: f = f0 + f1(P)
    A = 1e-3 * RNG.standard_normal((3, 3))
    P = A + A.T
    u = 0.02 * RNG.standard_normal(3)
    rho = 1.003
    f = O.feq(rho, u) + O.fone(P, u)
    tau = 0.7
    sig, uu = O.stress(f, tau)
    want = -(rho - 1) / 3 * np.eye(3) + (1 / (2 * tau) - 1) * P
    assert np.abs(sig - want).max() < 1e-16
    assert np.abs(uu - u).max() < 1e-15


def test_periodic_box_conservation_and_shift():
    shape = (6, 5, 7)
    rho, u = _fields(shape, 3)
    s = O.Sim(7, 5, 6, tau=0.6)
    s.init_fields(rho, u)
    f = s.f()
    xi, _ = O.lattice()
    m0 = f.sum()
    j0 = np.einsum("zyxi,ia->a", f, xi)
    s.fluid_step(60)
    f = s.f()
    assert abs(f.sum() - m0) < 1e-11
    assert np.abs(np.einsum("zyxi,ia->a", f, xi) - j0).max() < 1e-12
    # translation invariance: a shifted initial state gives the shifted solution bitwise
    s2 = O.Sim(7, 5, 6, tau=0.6)
    s2.init_fields(np.roll(rho, (1, 2, 3), axis=(0, 1, 2)), np.roll(u, (1, 2, 3), axis=(0, 1, 2)))
    s2.fluid_step(60)
    assert np.array_equal(s2.f(), np.roll(f, (1, 2, 3), axis=(0, 1, 2)))


def _fields(shape, seed):
    r = np.random.default_rng(seed)
    rho = 1 + 1e-3 * r.standard_normal(shape)
    u = 1e-2 * r.standard_normal(shape + (3,))
    return rho, u


def _tgv_rate(N, tau, steps):
    # 2-D shear-wave / Taylor-Green mode u_x = A sin(k y) in a periodic box
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / N
    shape = (2, N, N)
    y = np.arange(N)
    u = np.zeros(shape + (3,))
    x = np.arange(N)
    A = 1e-4
    u[..., 0] = A * np.sin(k * y)[None, :, None] * np.cos(k * x)[None, None, :]
    u[..., 1] = -A * np.cos(k * y)[None, :, None] * np.sin(k * x)[None, None, :]
    s = O.Sim(N, N, 2, tau=tau)
    s.init_fields(np.ones(shape), u)
    s.fluid_step(steps // 2)
    a1 = np.abs(s.velocity()[..., 0]).max()
    s.fluid_step(steps - steps // 2)
    a2 = np.abs(s.velocity()[..., 0]).max()
    rate = -math.log(a2 / a1) / (steps - steps // 2)
    return rate, 2 * nu * k * k


def test_taylor_green_decay_rate():
    errs = []
    for N in (16, 32):
        rate, want = _tgv_rate(N, 0.8, 200 if N == 16 else 400)
        errs.append(abs(rate / want - 1))
    assert errs[1] < 0.01
    assert errs[1] < errs[0]


@pytest.mark.parametrize("tau", [0.56, 0.65, 0.9])
def test_poiseuille_bgk_shift(tau):
    H = 32
    nu = (tau - 0.5) / 3.0
    g = 1e-6
    s = O.Sim(1, 1, H, tau=tau, bc_bottom=1, bc_top=1)
    z = np.arange(H)
    exact = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    u0 = np.zeros((H, 1, 1, 3))
    u0[:, 0, 0, 0] = exact
    s.init_fields(np.ones((H, 1, 1)), u0)
    h = np.zeros((H, 1, 1, 3))
    h[..., 0] = g
    s.set_force(h)
    tdiff = H * H / (math.pi ** 2 * nu)
    s.fluid_step(int(6 * tdiff))
    ux = s.velocity()[:, 0, 0, 0]
    err = np.sqrt(((ux - exact) ** 2).sum() / (exact ** 2).sum())
    assert err < 0.01, err


def test_poiseuille_literal_injects_tau_times_force():
    # the printed forcing (Eq. 15) adds tau*rho*h per step: the steady profile scales with tau
    tau, H, g = 0.65, 16, 1e-6
    nu = (tau - 0.5) / 3.0
    s = O.Sim(1, 1, H, tau=tau, bc_bottom=1, bc_top=1, force_scheme=1)
    z = np.arange(H)
    exact = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    s.init_fields()
    h = np.zeros((H, 1, 1, 3))
    h[..., 0] = g
    s.set_force(h)
    s.fluid_step(int(8 * H * H / (math.pi ** 2 * nu)))
    ux = s.velocity()[:, 0, 0, 0]
    ratio = ux.sum() / exact.sum()
    assert abs(ratio - tau) < 0.02


def test_pressure_top_ghost_is_rest_equilibrium_for_fluid_at_rest():
    s = O.Sim(4, 4, 6, tau=0.7, bc_bottom=1, bc_top=2, sponge=3)
    s.init_fields()
    s.fluid_step(5)
    xi, w = O.lattice()
    assert np.abs(s.f() - w).max() < 1e-15


def test_pressure_top_keeps_uniform_tangential_flow():
    # reading of the constant-pressure top (Sec. 2.5): ghost = f0(rho = 1, u of the
    # top plane).  A uniform tangential flow at rest density is then an exact fixed
    # point; a ghost at rest (u = 0) or a bounce-back top would shear it.
    nz, ny, nx = 8, 4, 5
    u = np.zeros((nz, ny, nx, 3))
    u[..., 0] = 0.03
    u[..., 1] = -0.01
    for top in (2, 1):
        s = O.Sim(nx, ny, nz, tau=0.7, bc_bottom=0, bc_top=top)
        s.init_fields(np.ones((nz, ny, nx)), u)
        s.fluid_step(20)
        dev = np.abs(s.velocity() - u).max()
        if top == 2:
            assert dev < 1e-15
        else:
            assert dev > 1e-4


def test_sponge_raises_viscosity_towards_the_top():
    # a shear wave u_x(y) decays faster inside the sponge (tau -> 1 at the top) than
    # below it; with tau0 = 1 the sponge changes nothing
    nz, ny, nx = 12, 16, 2
    y = np.arange(ny)
    u = np.zeros((nz, ny, nx, 3))
    u[..., 0] = 1e-3 * np.sin(2 * np.pi * y / ny)[None, :, None]
    s = O.Sim(nx, ny, nz, tau=0.55, bc_bottom=0, bc_top=2, sponge=6)
    s.init_fields(np.ones((nz, ny, nx)), u)
    s.fluid_step(30)
    amp = np.abs(s.velocity()[..., 0]).max(axis=(1, 2))
    assert amp[-1] < 0.8 * amp[0]
    s1 = O.Sim(nx, ny, nz, tau=1.0, bc_bottom=0, bc_top=2, sponge=6)
    s2 = O.Sim(nx, ny, nz, tau=1.0, bc_bottom=0, bc_top=2, sponge=0)
    for q in (s1, s2):
        q.init_fields(np.ones((nz, ny, nx)), u)
        q.fluid_step(10)
    assert np.array_equal(s1.velocity(), s2.velocity())


def test_sponge_profile_from_steady_shear_with_variable_viscosity():
    # The sponge of Sec. 2.5 raises the viscosity linearly to tau = 1 on the
    # top plane.  Steady plane Couette flow transmits one shear stress S through
    # every plane, so the velocity gradient is S / nu(z): the viscosity of each
    # plane is read off the steady profile, with S taken in the uniform part
    # below the sponge where nu = nu0 is known.  Every sponge plane must carry
    # nu(z) = (tau(z) - 1/2) / 3 with tau rising by (1 - tau0) / L per plane
    # from tau0 just below the sponge to 1 on the top plane (one plane of
    # shift is a 3-4 % change here; the centred differences of a smooth
    # profile are good to ~1e-3).
    nz, L, tau0, U = 40, 16, 0.8, 0.02
    z = np.arange(nz)
    # start near the steady state: u rising as the running integral of a rough
    # 1/nu guess (the linear profile below, doubled viscosity at the top);
    # what is left decays as exp(-nu0 (pi / H)^2 t), e^-7 over the run
    guess = 1.0 / np.where(z < nz - L, 1.0, 1.0 + (z - (nz - L) + 1) / L)
    prof = np.cumsum(guess) - 0.5 * guess
    u = np.zeros((nz, 2, 2, 3))
    u[..., 0] = (-U + 2 * U * prof / (prof[-1] + 0.5 * guess[-1]))[:, None, None]
    threads = O.get_threads()
    O.set_threads(2)
    try:
        s = O.Sim(2, 2, nz, tau0, bc_bottom=3, bc_top=3, sponge=L, uw_bottom=(-U, 0, 0), uw_top=(U, 0, 0))
        s.init_fields(None, u)
        s.fluid_step(12000)
        ux = s.velocity()[:, 0, 0, 0]
    finally:
        O.set_threads(threads)
    du = np.gradient(ux)  # centred differences inside
    nu0 = (tau0 - 0.5) / 3.0
    S = nu0 * np.mean(du[4:nz - L - 4])
    assert np.abs(du[4:nz - L - 4] * nu0 / S - 1.0).max() < 1e-4  # uniform stress below the sponge
    zs = np.arange(nz - L + 1, nz - 1)  # sponge planes with both neighbours inside it
    tau = tau0 + (1.0 - tau0) * (zs - (nz - L) + 1) / L
    nu_expected = (tau - 0.5) / 3.0
    nu_measured = S / du[zs]
    print("nu measured / expected per sponge plane:", np.round(nu_measured / nu_expected, 5))
    assert np.abs(nu_measured / nu_expected - 1.0).max() < 1e-2, nu_measured / nu_expected
    # and the profile is not a plane off either way
    for shift in (-1, 1):
        tau_s = tau0 + (1.0 - tau0) * (zs + shift - (nz - L) + 1) / L
        assert np.abs(nu_measured / ((tau_s - 0.5) / 3.0) - 1.0).max() > 2e-2


@pytest.mark.parametrize("u_bottom,u_top", [((0.0, 0.0, 0.0), (0.02, 0.0, 0.0)), ((0.0, -0.015, 0.0), (0.0, 0.015, 0.0))])
def test_moving_walls_couette_profile_and_shear_stress(u_bottom, u_top):
    # steady plane Couette flow between halfway-bounce-back walls at z = -1/2
    # and z = H - 1/2 moving in their planes: u(z) = u_b + (u_t - u_b)(z + 1/2)/H
    # (exact for the linear profile), and the shear stress nu (u_t - u_b)/H
    nz, tau = 16, 0.8
    s = O.Sim(4, 4, nz, tau, bc_bottom=3, bc_top=3, uw_bottom=u_bottom, uw_top=u_top)
    s.init_fields()
    s.fluid_step(10000)  # slowest mode decays as exp(-nu (pi / H)^2 t): e^-38
    u = s.velocity()
    ub, ut = np.array(u_bottom), np.array(u_top)
    z = np.arange(nz)
    ex = ub[None, :] + (ut - ub)[None, :] * ((z + 0.5) / nz)[:, None]
    scale = np.abs(ut - ub).max()
    assert np.abs(u - ex[:, None, None, :]).max() < 1e-10 * scale
    nu = (tau - 0.5) / 3.0
    sig = s.stress().reshape(nz, 4, 4, 3, 3)
    a = int(np.argmax(np.abs(ut - ub)))  # the sheared component
    assert np.abs(sig[:, :, :, a, 2] - nu * (ut - ub)[a] / nz).max() < 1e-10 * nu * scale / nz
