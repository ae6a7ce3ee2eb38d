"""Pins of the oracle's immersed-boundary parts: the Peskin kernel, transfer
operators, the multi-direct-forcing loop, and the surface-mesh properties."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_15115_gb300 import inputs as I

RNG = np.random.default_rng(77)


def test_peskin_closed_values():
    # Sec. 2.2 kernel at points where the square roots are exact
    assert O.peskin(0.0) == 0.5
    assert O.peskin(1.0) == 0.25
    assert O.peskin(2.0) == 0.0
    assert O.peskin(2.5) == 0.0
    assert abs(O.peskin(0.5) - (2 + math.sqrt(2)) / 8) < 1e-16
    assert abs(O.peskin(1.5) - (2 - math.sqrt(2)) / 8) < 1e-16
    assert O.peskin(-0.7) == O.peskin(0.7)


def test_peskin_moment_conditions():
    # the defining discrete conditions of the 4-point kernel (Peskin 2002):
    # sum w = 1, even and odd sums 1/2, first moment 0, sum w^2 = 3/8
    for r in RNG.uniform(0, 1, 50):
        js = np.arange(-3, 4)
        w = np.array([O.peskin(r - j) for j in js])
        assert abs(w.sum() - 1) < 1e-14
        assert abs(w[js % 2 == 0].sum() - 0.5) < 1e-14
        assert abs(((r - js) * w).sum()) < 1e-14
        assert abs((w * w).sum() - 3 / 8) < 1e-14


def _markers(n, shape):
    nz, ny, nx = shape
    return np.stack([RNG.uniform(2, nx - 3, n), RNG.uniform(2, ny - 3, n), RNG.uniform(2, nz - 3, n)], 1)


def test_interp_linear_field_exact_and_adjoint():
    shape = (12, 11, 10)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    field = np.stack([0.3 + 0.01 * x - 0.02 * y, 0.1 * z, 0.5 * x + 0.25 * y + 0.125 * z], -1)
    X = _markers(40, shape)
    per = (False, False, False)
    got = O.interp(field, X, per)
    want = np.stack([0.3 + 0.01 * X[:, 0] - 0.02 * X[:, 1], 0.1 * X[:, 2],
                     0.5 * X[:, 0] + 0.25 * X[:, 1] + 0.125 * X[:, 2]], -1)
    assert np.abs(got - want).max() < 1e-13
    # adjointness <I[u], h dS> = <u, S[h]> and total-force conservation
    u = RNG.standard_normal(shape + (3,))
    h = RNG.standard_normal((40, 3))
    dS = RNG.uniform(0.5, 1.5, 40)
    Iu = O.interp(u, X, per)
    Sh = O.spread(h, X, dS, shape, per)
    assert abs((Iu * h * dS[:, None]).sum() - (u * Sh).sum()) < 1e-12
    assert np.abs(Sh.reshape(-1, 3).sum(0) - (h * dS[:, None]).sum(0)).max() < 1e-12


def test_periodic_wrap_interp():
    shape = (8, 8, 8)
    u = RNG.standard_normal(shape + (3,))
    X = np.array([[0.3, 7.6, 4.2]])
    got = O.interp(u, X, (True, True, True))
    # same as interpolating in a rolled copy where the point is interior
    got2 = O.interp(np.roll(u, (0, -4, 4), axis=(0, 1, 2)), X + np.array([[4, -4, 0]]), (True, True, True))
    assert np.abs(got - got2).max() < 1e-14


def _phi_matrix(X, shape):
    # dense Phi[cell, k] = w(x-X) w(y-Y) w(z-Z) from the printed kernel, vectorised
    nz, ny, nx = shape
    def w(r):
        a = np.abs(r)
        out = np.zeros_like(a)
        m1 = a <= 1
        m2 = (a > 1) & (a <= 2)
        out[m1] = (3 - 2 * a[m1] + np.sqrt(1 + 4 * a[m1] - 4 * a[m1] ** 2)) / 8
        out[m2] = (5 - 2 * a[m2] - np.sqrt(np.maximum(0, -7 + 12 * a[m2] - 4 * a[m2] ** 2))) / 8
        return out
    wx = w(np.arange(nx)[:, None] - X[None, :, 0])
    wy = w(np.arange(ny)[:, None] - X[None, :, 1])
    wz = w(np.arange(nz)[:, None] - X[None, :, 2])
    return (wz[:, None, None, :] * wy[None, :, None, :] * wx[None, None, :, :]).reshape(-1, X.shape[0])


def test_ibm_loop_equals_neumann_series():
    # IBM steps l=0..4, n=4 cycles: h^(3) = sum_{j=0..3} (I - A)^j r0 with A = I o S,
    # r0 = U - I[u*]; h_imm = S[h^(3)]  (algebra of Sec. 2.2, A built densely here)
    shape = (14, 14, 14)
    V, T = I.icosphere(2, 3.0)
    X = V + 7.0 + RNG.uniform(-0.3, 0.3, 3)
    mp = O.mesh_props(V, T)
    dS = mp["dS"]
    ustar = 0.01 * RNG.standard_normal(shape + (3,))
    U = 0.01 * RNG.standard_normal((X.shape[0], 3))
    himm, hl = O.ibm(ustar, X, U, dS, 4, (False, False, False))
    Phi = _phi_matrix(X, shape)
    A = Phi.T @ (Phi * dS[None, :])
    r0 = U - Phi.T @ ustar.reshape(-1, 3)
    M = np.eye(A.shape[0]) - A
    h = r0.copy()
    term = r0.copy()
    for _ in range(3):
        term = M @ term
        h += term
    assert np.abs(hl - h).max() < 1e-12
    assert np.abs(himm.reshape(-1, 3) - Phi @ (h * dS[:, None])).max() < 1e-12


def _cube():
    V = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], dtype=float)
    # outward CCW faces
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    T = []
    for a, b, c, d in quads:
        T += [(a, b, c), (a, c, d)]
    return V, np.array(T, dtype=np.int32)


def test_mass_properties_cube_and_tetrahedron():
    V, T = _cube()
    p = O.mesh_props(V, T)
    assert abs(p["volume"] - 1) < 1e-15
    assert np.abs(p["com"] - 0.5).max() < 1e-15
    assert np.abs(p["J_over_m"] - np.eye(3) / 6).max() < 1e-15
    assert abs(p["area"] - 6) < 1e-14 and abs(p["dS"].sum() - 6) < 1e-14
    # unit simplex: Dirichlet integrals int x^2 = 1/60, int xy = 1/120, V = 1/6, c = 1/4
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    T = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], dtype=np.int32)
    p = O.mesh_props(V, T)
    assert abs(p["volume"] - 1 / 6) < 1e-16
    assert np.abs(p["com"] - 0.25).max() < 1e-16
    Sxx, Sxy = 1 / 60 - (1 / 6) / 16, 1 / 120 - (1 / 6) / 16
    Jxx = (3 * Sxx - Sxx) * 6
    Jxy = -Sxy * 6
    want = np.full((3, 3), Jxy)
    np.fill_diagonal(want, Jxx)
    assert np.abs(p["J_over_m"] - want).max() < 1e-15


def test_mass_properties_ellipsoid_second_order():
    a, b, c = 8.0, 4.0, 3.0
    exact = np.diag([b * b + c * c, a * a + c * c, a * a + b * b]) / 5
    errs = []
    for n in (6, 12):
        V, T = I.ellipsoid(n, (a, b, c))
        p = O.mesh_props(V, T)
        errs.append(np.abs(p["J_over_m"] - exact).max() / exact.max())
        assert np.abs(p["com"]).max() < 1e-12
    assert errs[1] < 0.01
    assert 3.0 < errs[0] / errs[1] < 5.0  # O(h^2)


def test_sphere_normals_radial_and_area():
    V, T = I.icosphere(5, 4.0)
    p = O.mesh_props(V, T)
    radial = V / np.linalg.norm(V, axis=1, keepdims=True)
    assert np.einsum("ij,ij->i", p["normals"], radial).min() > 0.999
    assert abs(p["dS"].sum() - p["area"]) < 1e-13 * p["area"]


def test_open_mesh_rejected():
    V, T = I.icosphere(2, 1.0)
    with pytest.raises(ValueError):
        O.mesh_props(V, T[1:])
    with pytest.raises(ValueError):
        O.mesh_props(V, T[:, ::-1])  # inward orientation gives negative volume


@pytest.mark.parametrize("ncycles", [1, 3, 4])
def test_warm_started_ibm_cycles_equal_their_closed_form(ncycles):
    # predictor option: the cycles start from a given h0 instead of U - I[u*];
    # with no early stop (eps 0), C cycles give
    # h_C = (I - A)^C h0 + sum_{j<C} (I - A)^j r0, r0 = U - I[u*], A = I o S
    # (built densely here), and h_imm = S[h_C]
    shape = (14, 14, 14)
    V, T = I.icosphere(2, 3.0)
    X = V + 7.0 + RNG.uniform(-0.3, 0.3, 3)
    dS = O.mesh_props(V, T)["dS"]
    ustar = 0.01 * RNG.standard_normal(shape + (3,))
    U = 0.01 * RNG.standard_normal((X.shape[0], 3))
    h0 = 0.01 * RNG.standard_normal((X.shape[0], 3))
    himm, h, run = O.ibm_warm(ustar, X, U, dS, h0, ncycles, 0.0, (False, False, False))
    assert run == ncycles
    Phi = _phi_matrix(X, shape)
    A = Phi.T @ (Phi * dS[None, :])
    r0 = U - Phi.T @ ustar.reshape(-1, 3)
    M = np.eye(A.shape[0]) - A
    want = h0.copy()
    for _ in range(ncycles):
        want = M @ want + r0
    assert np.abs(h - want).max() < 1e-12
    assert np.abs(himm.reshape(-1, 3) - Phi @ (h * dS[:, None])).max() < 1e-12
    # a slip tolerance above the first cycle's residual stops after one cycle
    res1 = np.abs(r0 - A @ h0).max()
    _, h1, run1 = O.ibm_warm(ustar, X, U, dS, h0, 4, 2.0 * res1, (False, False, False))
    assert run1 == 1
    assert np.abs(h1 - (M @ h0 + r0)).max() < 1e-12
