"""Shared set-up of GPU-vs-oracle parity cases: the same seeded inputs are
handed to the CUDA path (through the C ABI) and to the oracle."""
import numpy as np

from oracle import oracle as O
from paper_2408_15115_gb300 import inputs as I

# velocity parity bar for FP32 storage (max-norm relative, after 100 steps)
TOL_U_F32 = 1e-5


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def oracle_velocity(sim):
    return sim.velocity()  # (nz, ny, nx, 3)


def gpu_velocity(t):
    m = t.macro().cpu().numpy().astype(np.float64)  # (4, nz, ny, nx)
    return np.moveaxis(m[1:], 0, -1), m[0]


def make_pair(nx, ny, nz, nu, bc, kappa=1.0, g=(0, 0, 0), sponge=0, slide=0, anchor=0.25, storage="f32",
              flags=None, fields=None, particle=None, walls=None, reinject=None, predictor=None):
    """Build a (Turret, oracle Sim) pair with identical configuration.

    bc = (bc_x, bc_y, bc_bottom, bc_top); fields = (rho, u) or None;
    particle = (verts, tris, r0, v0, w0) or None; walls = (u_bottom, u_top)
    for moving walls (bc 3) or None; reinject = (trigger, target, below,
    above) for the re-injection copy or None; predictor = (warm, eps) for the
    linear-extrapolation predictor with predicted marker velocities (and
    warm-started cycles when warm) or None."""
    from paper_2408_15115_gb300 import turret as T
    flags = dict(flags or {})
    tau = 3 * nu + 0.5
    t = T.Turret(nx, ny, nz, nu, kappa, g, *bc, sponge=sponge, slide=slide, anchor_frac=anchor, storage=storage,
                 flags=flags or None)
    s = O.Sim(nx, ny, nz, tau, *bc, sponge=sponge, slide=slide, anchor_frac=anchor,
              force_scheme=flags.get("force_scheme", 0), rot_form=flags.get("rot_form", 0),
              gravity=flags.get("gravity", 0), renorm=flags.get("renorm_orientation", 0),
              ibm_cycles=flags.get("ibm_cycles", 4), kappa=kappa, g=g,
              fixed_position=flags.get("fixed_position", 0),
              uw_bottom=walls[0] if walls else (0, 0, 0), uw_top=walls[1] if walls else (0, 0, 0),
              reinject=reinject or (0, 0, 0, 0), force_eval=flags.get("force_eval", 0),
              predictor=1 if predictor else 0, pred_warm=int(predictor[0]) if predictor else 0,
              pred_eps=float(predictor[1]) if predictor else 0.0)
    if predictor is not None:
        t.set_predictor("linear", warm=bool(predictor[0]), velocity=True, slip_eps=float(predictor[1]))
    if reinject is not None:
        t.set_reinjection(*reinject)
    if walls is not None:
        t.set_wall_velocity(*walls)
    if fields is not None:
        rho, u = fields
        t.set_fields(rho, u)
        s.init_fields(rho, u)
    else:
        s.init_fields()
    if particle is not None:
        V, Tr, r0, v0, w0 = particle
        t.load_surface(V, Tr, r0, v0, w0)
        s.load_particle(V, Tr, r0, v0, w0)
    return t, s


def sphere_case(n=5, d=8.0):
    return I.sphere(n, d)


def k_cyl(lam):
    """Haberman-Sayre wall factor K(d / D) of the Stokes drag of a sphere on the
    axis of a long cylinder, from tests/golden/haberman_sayre_1958_wall_factor.txt."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "haberman_sayre_1958_wall_factor.txt")
    k = 0.0
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            n, c = line.split()
            k += float(c) * lam ** int(n)
    return k

