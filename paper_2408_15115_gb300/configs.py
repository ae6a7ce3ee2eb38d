"""Synthetic workloads in lattice units (dx = dt = 1) for the settling cases.

Each workload keeps the paper's set-up (Sec. 2.5 and Table 2): a window that
is periodic laterally, no-slip at the bottom, constant pressure with a sponge
at the top, the time step normalised so that the terminal velocity is about
0.02 (Sec. 3 opening), gravity along -z.  Where only a Reynolds number is
given, g follows from the Clift-Gauvin drag curve (Eq. 28) for the
volume-equivalent sphere with the buoyancy-reduced weight:
(kappa - 1) V g = C_D(Re) pi d^2 v^2 / 8.
"""
import math

import numpy as np

from . import inputs as I
from .analysis import cg71_cd  # Clift & Gauvin (1971) drag coefficient, Eq. 28


def gravity_for(re, d, nu, kappa):
    """|g| (lattice units) that makes a sphere of diameter d settle at Reynolds number re."""
    v = re * nu / d
    return 3.0 * cg71_cd(re) * v * v / (4.0 * d * (kappa - 1.0))


def sphere_box():
    """32 x 32 x 64 closed box, sphere d = 8 (252 markers), nu 0.05, kappa 2.5, g 1e-5 (Re ~ 0.2)."""
    V, T = I.sphere(5, 8.0)
    return dict(name="sphere_32x32x64_closed", nx=32, ny=32, nz=64, nu=0.05, kappa=2.5, g=(0.0, 0.0, -1e-5),
                bc=(1, 1, 1, 1), sponge=0, slide=0, anchor=0.25, storage="f32", verts=V, tris=T,
                r0=(15.5, 15.5, 44.0))


def prolate_turret(storage="f32"):
    """96 x 96 x 192 sliding turret window, prolate spheroid 16:8:8 (812 markers)
    tilted 30 degrees about x, nu 0.02, kappa 2, g from Eq. 28 at Re ~ 10."""
    V, T = I.ellipsoid(9, (4.0, 8.0, 4.0))  # major axis (16) along y
    V = I.rotate(V, "x", 30.0)
    d_eq = (6.0 * (4.0 / 3.0) * math.pi * 4.0 * 8.0 * 4.0 / math.pi) ** (1.0 / 3.0)
    nu, kappa = 0.02, 2.0
    g = gravity_for(10.0, d_eq, nu, kappa)
    return dict(name="prolate_96x96x192_turret", nx=96, ny=96, nz=192, nu=nu, kappa=kappa, g=(0.0, 0.0, -g),
                bc=(0, 0, 1, 2), sponge=15, slide=1, anchor=0.25, storage=storage, verts=V, tris=T,
                r0=(47.5, 47.5, 48.0), d_eq=d_eq)


def irregular_turret(storage="f16"):
    """192 x 192 x 384 window, spherical-harmonic particle d_eq = 24 (3612 markers), Re ~ 200."""
    V, T = I.sh_particle(19, 24.0, seed=3)
    nu, kappa = 0.02 * 24.0 / 200.0, 2.0
    g = gravity_for(200.0, 24.0, nu, kappa)
    return dict(name="irregular_192x192x384_turret", nx=192, ny=192, nz=384, nu=nu, kappa=kappa, g=(0.0, 0.0, -g),
                bc=(0, 0, 1, 2), sponge=30, slide=1, anchor=0.25, storage=storage, verts=V, tris=T,
                r0=(95.5, 95.5, 96.0), d_eq=24.0)


def irregular_large(storage="f16"):
    """256 x 256 x 512 window, spherical-harmonic particle d_eq = 32 (6252 markers), Re ~ 1000."""
    V, T = I.sh_particle(25, 32.0, seed=5)
    nu, kappa = 0.02 * 32.0 / 1000.0, 2.0
    g = gravity_for(1000.0, 32.0, nu, kappa)
    return dict(name="irregular_256x256x512_turret", nx=256, ny=256, nz=512, nu=nu, kappa=kappa, g=(0.0, 0.0, -g),
                bc=(0, 0, 1, 2), sponge=40, slide=1, anchor=0.25, storage=storage, verts=V, tris=T,
                r0=(127.5, 127.5, 128.0), d_eq=32.0)


WORKLOADS = {"sphere_box": sphere_box, "prolate_turret": prolate_turret, "irregular_turret": irregular_turret,
             "irregular_large": irregular_large}


def make_turret(cfg, **kw):
    from .turret import Turret
    t = Turret(cfg["nx"], cfg["ny"], cfg["nz"], cfg["nu"], cfg["kappa"], cfg["g"], *cfg["bc"], sponge=cfg["sponge"],
               slide=cfg["slide"], anchor_frac=cfg["anchor"], storage=cfg["storage"], **kw)
    return t


ENSEMBLE_SHAPES = ("sphere", "oblate", "prolate", "irregular")
ENSEMBLE_WINDOWS = ((64, 64, 64), (96, 96, 192), (128, 128, 256))


def _freq_for(r_max, spacing=0.9):
    """Icosphere frequency giving marker spacing about ``spacing`` on a surface
    whose largest radius is r_max (the geodesic edge is about 1.2 r / n)."""
    return max(4, int(math.ceil(1.2 * r_max / spacing)))


def ensemble_member(shape, d, re, window, storage, seed, kappa=2.0):
    """One settling run of the ensemble: a particle of volume-equivalent
    diameter d (sphere, oblate 1:2, prolate 2:1 or spherical-harmonic
    irregular), nu = 0.02 d / Re, g from Eq. 28, in a sliding turret window."""
    rng = np.random.default_rng(seed)
    R = 0.5 * d
    if shape == "sphere":
        V, T = I.sphere(_freq_for(R), d)
    elif shape == "oblate":
        a = R * 2.0 ** (1.0 / 3.0)  # semi-axes (a, a, a/2): volume of the sphere of radius R
        V, T = I.ellipsoid(_freq_for(a), (a, a, 0.5 * a))
    elif shape == "prolate":
        b = R / 2.0 ** (1.0 / 3.0)  # semi-axes (2b, b, b)
        V, T = I.ellipsoid(_freq_for(2.0 * b), (2.0 * b, b, b))
    else:
        V, T = I.sh_particle(_freq_for(1.2 * R), d, seed=int(rng.integers(1 << 30)))
    if shape != "sphere":
        V = I.rotate(I.rotate(V, "x", float(rng.uniform(0.0, 45.0))), "z", float(rng.uniform(0.0, 90.0)))
    nx, ny, nz = window
    nu = 0.02 * d / re
    g = gravity_for(re, d, nu, kappa)
    return dict(name="%s_d%.1f_re%.1f_%dx%dx%d" % (shape, d, re, nx, ny, nz), nx=nx, ny=ny, nz=nz, nu=nu,
                kappa=kappa, g=(0.0, 0.0, -g), bc=(0, 0, 1, 2), sponge=int(round(0.08 * nz)), slide=1,
                anchor=0.25, storage=storage, verts=V, tris=T,
                r0=(0.5 * nx - 0.5, 0.5 * ny - 0.5, 0.25 * nz + 0.5), d_eq=d, re=re, shape=shape)


def ensemble(n_runs=64, seed=4, storage="alternate", d_range=(8.0, 24.0), re_range=(1.0, 100.0)):
    """Independent settling runs drawn by seed: shape uniform over
    ENSEMBLE_SHAPES, d ~ U(d_range), Re log-uniform over re_range, window the
    smallest of ENSEMBLE_WINDOWS at least 4 d wide; storage 'alternate'
    (FP32, FP16, FP32, ...) or one storage name for every run."""
    rng = np.random.default_rng(seed)
    runs = []
    for k in range(n_runs):
        shape = ENSEMBLE_SHAPES[int(rng.integers(len(ENSEMBLE_SHAPES)))]
        d = float(rng.uniform(*d_range))
        re = float(math.exp(rng.uniform(math.log(re_range[0]), math.log(re_range[1]))))
        window = next(w for w in ENSEMBLE_WINDOWS if w[0] >= 4.0 * d or w is ENSEMBLE_WINDOWS[-1])
        st = ("f32" if k % 2 == 0 else "f16") if storage == "alternate" else storage
        runs.append(ensemble_member(shape, d, re, window, st, seed=int(rng.integers(1 << 30))))
    return runs


def load_ensemble(cfgs, **kw):
    """Turret objects with loaded surfaces for a list of ensemble configurations."""
    out = []
    for c in cfgs:
        t = make_turret(c, **kw)
        t.load_surface(c["verts"], c["tris"], c["r0"])
        out.append(t)
    return out
