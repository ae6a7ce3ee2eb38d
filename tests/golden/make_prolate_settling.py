"""Writes the long-horizon settling trajectory of the prolate turret workload
computed by the FP64 oracle, the stored expected values of the full-run GPU
parity test (drag, settling velocity and orientation over thousands of steps).

Workload: the 96 x 96 x 192 sliding turret window (periodic sides, no-slip
bottom, constant-pressure top with a 15-plane sponge), a prolate spheroid
16:8:8 (icosphere frequency 9, 812 markers) tilted 30 degrees about x,
nu = 0.02, kappa = 2, g from the Clift-Gauvin drag curve (Eq. 28) at Re ~ 10,
released from rest.  Every SAMPLE steps one row: step, window origin z, centre
r (window coordinates), v, w, F, Fp, T and the orientation matrix d (rows:
the body axes in the lab frame, Sec. 2.3).

Only the oracle and the seeded input generators are called.  Usage:

    python tests/golden/make_prolate_settling.py STEPS FORCE_EVAL THREADS

force_eval 0: stress integrated on the offset surface X + 2n (the library's
default); 1: at the markers, as printed at the end of Sec. 2.2.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2408_15115_gb300 import configs  # noqa: E402

SAMPLE = 10
COLUMNS = ("step origin_z rx ry rz vx vy vz wx wy wz Fx Fy Fz Fpx Fpy Fpz Tx Ty Tz "
           "d00 d01 d02 d10 d11 d12 d20 d21 d22")


def path_for(force_eval):
    return os.path.join(HERE, "prolate_96x96x192_settling_fe%d.txt" % force_eval)


def main():
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 3000
    force_eval = int(sys.argv[2]) if len(sys.argv) > 2 else 0
    threads = int(sys.argv[3]) if len(sys.argv) > 3 else (os.cpu_count() or 1)
    O.set_threads(threads)
    cfg = configs.prolate_turret()
    s = O.Sim(cfg["nx"], cfg["ny"], cfg["nz"], 3 * cfg["nu"] + 0.5, *cfg["bc"], sponge=cfg["sponge"],
              slide=cfg["slide"], anchor_frac=cfg["anchor"], kappa=cfg["kappa"], g=cfg["g"], force_eval=force_eval)
    s.init_fields()
    s.load_particle(cfg["verts"], cfg["tris"], cfg["r0"])
    rows = []
    t0 = time.time()
    for k in range(steps // SAMPLE):
        s.step(SAMPLE)
        st = s.state()
        rows.append(np.concatenate([[st["step"], st["origin"][2]], st["r"], st["v"], st["w"], st["F"], st["Fp"],
                                    st["T"], st["d"].ravel()]))
        if (k + 1) % 50 == 0:
            print("step %d  %.0f s  vz %.6e  Fz %.6e" % (st["step"], time.time() - t0, st["v"][2], st["F"][2]),
                  flush=True)
    head = ("prolate 16:8:8 tilted 30 deg, 96x96x192 sliding turret window, nu 0.02, kappa 2, g %.10e, "
            "FP64 oracle, force_eval %d, %d steps from rest, one row every %d steps\n%s"
            % (-cfg["g"][2], force_eval, steps, SAMPLE, COLUMNS))
    tmp = path_for(force_eval) + ".tmp"
    np.savetxt(tmp, np.array(rows), fmt="%.17g", header=head)
    os.replace(tmp, path_for(force_eval))
    print("wrote", path_for(force_eval))


if __name__ == "__main__":
    main()
