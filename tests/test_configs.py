"""The seeded workload recipes (host logic, no GPU): the 64-run settling
ensemble of the batched benchmark and the single-particle workloads."""
import math

import numpy as np

from paper_2408_15115_gb300 import configs
from paper_2408_15115_gb300.analysis import cg71_terminal_velocity


def _mesh_volume(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


def test_ensemble_recipe_seed_4():
    # shape uniform over four families, d ~ U[8, 24], Re log-uniform on [1, 100],
    # the smallest window at least 4 d wide, storage alternating FP32 / FP16;
    # the seed-4 draw is the benchmark's: 27 windows of 64^3 and 37 of
    # 96 x 96 x 192, 72,548,352 cells and 145,828 markers
    runs = configs.ensemble(64, seed=4)
    windows = [(c["nx"], c["ny"], c["nz"]) for c in runs]
    assert windows.count((64, 64, 64)) == 27 and windows.count((96, 96, 192)) == 37
    assert sum(c["nx"] * c["ny"] * c["nz"] for c in runs) == 72_548_352
    assert sum(len(c["verts"]) for c in runs) == 145_828
    assert {c["shape"] for c in runs} == set(configs.ENSEMBLE_SHAPES)
    assert [c["storage"] for c in runs] == ["f32", "f16"] * 32
    for c in runs:
        assert 8.0 <= c["d_eq"] <= 24.0 and 1.0 <= c["re"] <= 100.0
        assert c["nx"] >= 4.0 * c["d_eq"]
        assert abs(c["nu"] - 0.02 * c["d_eq"] / c["re"]) < 1e-15
        # the particle has the volume of the sphere of diameter d
        vol = _mesh_volume(np.asarray(c["verts"]), np.asarray(c["tris"]))
        assert abs(vol / (math.pi * c["d_eq"] ** 3 / 6.0) - 1.0) < 0.02, (c["name"], vol)
        # g makes that sphere settle at Re by the drag curve of Eq. 28
        v = cg71_terminal_velocity(c["d_eq"], c["nu"], c["kappa"], -c["g"][2])
        assert abs(v * c["d_eq"] / c["nu"] / c["re"] - 1.0) < 1e-6
    # a draw is reproducible
    again = configs.ensemble(64, seed=4)
    assert all(np.array_equal(a["verts"], b["verts"]) and a["g"] == b["g"] for a, b in zip(runs, again))


def test_prolate_workload():
    # the benchmark's single window: 96 x 96 x 192, prolate 16:8:8 spheroid of
    # 812 markers, Re ~ 10 by Eq. 28 for the volume-equivalent sphere
    c = configs.prolate_turret()
    assert (c["nx"], c["ny"], c["nz"]) == (96, 96, 192) and len(c["verts"]) == 812
    d = c["d_eq"]
    assert abs(d - (16.0 * 8.0 * 8.0) ** (1.0 / 3.0)) < 1e-12
    v = cg71_terminal_velocity(d, c["nu"], c["kappa"], -c["g"][2])
    assert abs(v * d / c["nu"] - 10.0) < 1e-5
