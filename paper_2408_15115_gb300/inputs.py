"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle's.

This module holds no arithmetic of the method itself: it only makes shapes
(triangulated surfaces) and random initial fields, from fixed seeds.  Surface
meshes follow the particle families of the paper's validation cases (spheres,
spheroids, an irregular lapilli-like particle, Sec. 3); the scanned lapilli mesh
is not public, so a sphere with random real spherical-harmonic bumps stands in
for it.  Mesh vertices become the Lagrangian markers (Sec. 2.2).
"""
import math

import numpy as np


# --------------------------------------------------------------------------
# Geodesic icosphere (class I, frequency n): 10 n^2 + 2 vertices, 20 n^2 faces.

def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * phi))
            v.append((s1, s2 * phi, 0.0))
            v.append((s2 * phi, 0.0, s1))
    v = np.array(v)
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                if all(abs(np.linalg.norm(v[a] - v[b]) - 2.0) < 1e-9 for a, b in ((i, j), (j, k), (i, k))):
                    a, b, c = v[i], v[j], v[k]
                    if np.dot(np.cross(b - a, c - a), a + b + c) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    assert len(faces) == 20
    return v / np.linalg.norm(v, axis=1, keepdims=True), faces


def icosphere(n, radius=1.0):
    """Unit-sphere geodesic mesh of frequency n scaled to ``radius``.

    Returns (verts float64 [10n^2+2, 3], tris int32 [20n^2, 3]); triangles are
    counter-clockwise seen from outside."""
    base, faces = _icosahedron()
    verts, index = [], {}

    def vid(p):
        p = p / np.linalg.norm(p)
        key = tuple(np.round(p, 9))
        if key not in index:
            index[key] = len(verts)
            verts.append(p)
        return index[key]

    tris = []
    for (ia, ib, ic) in faces:
        A, B, Cc = base[ia], base[ib], base[ic]
        grid = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                grid[(i, j)] = vid(A + (B - A) * (i / n) + (Cc - A) * (j / n))
        for i in range(n):
            for j in range(n - i):
                tris.append((grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]))
                if i + j + 1 < n:
                    tris.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    V = np.array(verts) * radius
    T = np.array(tris, dtype=np.int32)
    assert V.shape[0] == 10 * n * n + 2 and T.shape[0] == 20 * n * n
    return V, T


def ellipsoid(n, semi_axes):
    """Icosphere of frequency n mapped onto an ellipsoid with semi-axes (a, b, c) along x, y, z."""
    V, T = icosphere(n, 1.0)
    return V * np.asarray(semi_axes, dtype=np.float64)[None, :], T


def rotate(verts, axis, angle_deg):
    """Rotate vertices by ``angle_deg`` about the coordinate axis 'x', 'y' or 'z'."""
    a = math.radians(angle_deg)
    c, s = math.cos(a), math.sin(a)
    R = {"x": [[1, 0, 0], [0, c, -s], [0, s, c]],
         "y": [[c, 0, s], [0, 1, 0], [-s, 0, c]],
         "z": [[c, -s, 0], [s, c, 0], [0, 0, 1]]}[axis]
    return verts @ np.array(R).T


def _mesh_volume(V, T):
    # shape normalisation only (scales a generated surface to a target size)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def _real_sh(lmax, theta, phi):
    """Real spherical harmonics up to lmax (l >= 1) at polar angle theta, azimuth phi."""
    x = np.cos(theta)
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    out = []
    # associated Legendre P_l^m(x) by the standard upward recurrences
    P = {}
    P[(0, 0)] = np.ones_like(x)
    for m in range(0, lmax + 1):
        if m > 0:
            P[(m, m)] = -(2 * m - 1) * sx * P[(m - 1, m - 1)]
        if m + 1 <= lmax:
            P[(m + 1, m)] = (2 * m + 1) * x * P[(m, m)]
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(norm * P[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2) * norm * P[(l, am)] * np.cos(am * phi))
            else:
                out.append(math.sqrt(2) * norm * P[(l, am)] * np.sin(am * phi))
    return np.stack(out, axis=0)


def sh_particle(n, d_eq, seed, amplitude=0.2, lmax=6):
    """Irregular closed surface: a frequency-n icosphere whose radius is
    perturbed by real spherical harmonics 1 <= l <= lmax with N(0,1) seeded
    coefficients, scaled so that max |dr|/R = amplitude on the vertices, then
    scaled to the volume-equivalent diameter d_eq and centred on the vertex mean."""
    V, T = icosphere(n, 1.0)
    rng = np.random.default_rng(seed)
    theta = np.arccos(np.clip(V[:, 2], -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    Y = _real_sh(lmax, theta, phi)
    coef = rng.standard_normal(Y.shape[0])
    dr = coef @ Y
    dr *= amplitude / np.max(np.abs(dr))
    V = V * (1.0 + dr)[:, None]
    vol = _mesh_volume(V, T)
    target = math.pi * d_eq ** 3 / 6.0
    V *= (target / vol) ** (1.0 / 3.0)
    V -= V.mean(axis=0, keepdims=True)
    return V, T


def sphere(n, d):
    return icosphere(n, 0.5 * d)


# --------------------------------------------------------------------------
# Smooth random initial fields (Fourier modes with integer wave numbers).

def smooth_field(shape, ncomp, amplitude, kmax, seed):
    """Sum of random Fourier modes with |k_a| <= kmax on an (nz, ny, nx) grid,
    returned as float64 (nz, ny, nx, ncomp), scaled to max |value| = amplitude."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros(shape + (ncomp,))
    for c in range(ncomp):
        acc = np.zeros(shape)
        for _ in range(12):
            k = rng.integers(-kmax, kmax + 1, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.standard_normal()
            acc += a * np.cos(2 * math.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + ph)
        out[..., c] = acc
    m = np.max(np.abs(out))
    if m > 0:
        out *= amplitude / m
    return out


def random_state(shape, u_amp=0.01, rho_amp=0.001, kmax=4, seed=1):
    """(rho, u) for a seeded smooth perturbed initial state: rho = 1 + drho."""
    u = smooth_field(shape, 3, u_amp, kmax, seed)
    drho = smooth_field(shape, 1, rho_amp, kmax, seed + 1000)[..., 0]
    return 1.0 + drho, u


# --------------------------------------------------------------------------
# Seeded initial weights of the force/torque surrogate network (34 -> 3 x 128
# -> 6, flat layout W1 b1 W2 b2 W3 b3 W4 b4): normal weights with variance
# 2 / fan_in (He et al. 2015), zero biases, returned as float64.

MLP_LAYERS = ((128, 34), (128, 128), (128, 128), (6, 128))


def mlp_init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for n_out, n_in in MLP_LAYERS:
        parts.append(rng.standard_normal(n_out * n_in) * math.sqrt(2.0 / n_in))
        parts.append(np.zeros(n_out))
    return np.concatenate(parts)
